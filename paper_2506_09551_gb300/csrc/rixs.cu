// The whole RIXS map (Eqs. 1-2) and the sector maps O2 = c^dag_{j,up},
// O1 = c_{j,up}.
//
// Pipeline of msb_rixs_map:
//   1. H on (n_up, n_dn) and H' = H - Uc (n_{j,up} + n_{j,dn}) on (n_up+1, n_dn).
//   2. |G>, E_G: FP64 Lanczos (unless the caller passes G).
//   3. E = O2 |G>.
//   4. One multi-shift solve (H' - E_G - i Gamma - w_seed - s_k) x_k = E with
//      s_k = w_in[k] - w_seed: x_k = Psi(w_in[k]) (Eq. 2, App. C).  Only the
//      components that O1 reads are carried per shift (the per-shift update is
//      elementwise, so the others are never needed): the rows u' of the
//      intermediate sector with site j occupied by the up electron.
//   5. phi_k = O1 Psi_k (Eq. 1).
//   6. Batched Lanczos continued fraction of H for every phi_k (Eq. 1).
#include <chrono>
#include <memory>
#include <cmath>
#include <vector>

#include "kernels.cuh"
#include "msbicg_impl.cuh"
#include "profile.cuh"

namespace msb {

// y[dst_row, d] = sign * x[src_row, d] for every column; map entry
// (src_row << 1) | neg, or -1 for a zero row.  Src real (double) or complex.
template <typename VS, typename VD>
__global__ void __launch_bounds__(256) k_rowmap(const VS* __restrict__ x, VD* __restrict__ y,
                                                const int32_t* __restrict__ map, int64_t rows_dst, int64_t Ddn,
                                                int64_t ld_x, int64_t ld_y) {
    const int64_t n = rows_dst * Ddn;
    const VS* __restrict__ xc = x + int64_t(blockIdx.y) * ld_x;
    VD* __restrict__ yc = y + int64_t(blockIdx.y) * ld_y;
    for (int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; s < n; s += int64_t(gridDim.x) * blockDim.x) {
        const int64_t row = s / Ddn, d = s - row * Ddn;
        const int32_t m = __ldg(map + row);
        VD out = vzero(VD{});
        if (m >= 0) {
            const VS v = xc[int64_t(m >> 1) * Ddn + d];
            if constexpr (is_cplx_v<VS>) {
                out = mk(scalar_t<VD>(v.x), scalar_t<VD>(v.y));
            } else {
                out = mk(scalar_t<VD>(v), scalar_t<VD>(0));
            }
            if (m & 1) out = vsub(vzero(VD{}), out);
        }
        yc[s] = out;
    }
}

static std::vector<int32_t> rank_table(const std::vector<uint32_t>& st, int L) {
    std::vector<int32_t> r(size_t(1) << L, -1);
    for (size_t i = 0; i < st.size(); ++i) r[st[i]] = int32_t(i);
    return r;
}

static inline int jw_sign_below(uint32_t u, int j) { return __builtin_popcount(u & ((1u << j) - 1u)) & 1; }

// Row map of c^dag_{j,up}: dst rows = up states with n+1 electrons.
static std::vector<int32_t> cdag_rowmap(int L, int n_up, int j) {
    auto src = sector_states(L, n_up), dst = sector_states(L, n_up + 1);
    auto rs = rank_table(src, L);
    std::vector<int32_t> m(dst.size(), -1);
    for (size_t r = 0; r < dst.size(); ++r) {
        const uint32_t u = dst[r];
        if (!((u >> j) & 1u)) continue;
        const uint32_t v = u ^ (1u << j);
        m[r] = (rs[v] << 1) | jw_sign_below(v, j);
    }
    return m;
}

// Row map of c_{j,up}: dst rows = up states with n electrons, src n+1.
static std::vector<int32_t> c_rowmap(int L, int n_up, int j) {
    auto dst = sector_states(L, n_up), src = sector_states(L, n_up + 1);
    auto rs = rank_table(src, L);
    std::vector<int32_t> m(dst.size(), -1);
    for (size_t r = 0; r < dst.size(); ++r) {
        const uint32_t u = dst[r];
        if ((u >> j) & 1u) continue;
        const uint32_t v = u | (1u << j);
        m[r] = (rs[v] << 1) | jw_sign_below(u, j);
    }
    return m;
}

template <typename VS, typename VD>
static void launch_rowmap(const VS* x, VD* y, const std::vector<int32_t>& map, int64_t Ddn, int64_t ld_x, int64_t ld_y,
                          int nvec, cudaStream_t st, int64_t& launches) {
    DevBuf<int32_t> dmap(map.size());
    dmap.upload(map.data(), map.size(), st);
    const int64_t n = int64_t(map.size()) * Ddn;
    {
        ProfScope ps("sector_map", st, double(nvec) * n * (sizeof(VS) + sizeof(VD)), 0);
        k_rowmap<VS, VD><<<dim3(grid_for(n, 256, 8), nvec), 256, 0, st>>>(x, y, dmap.p, int64_t(map.size()), Ddn,
                                                                           ld_x, ld_y);
    }
    MSB_LAUNCH_CHECK();
    MSB_CUDA(cudaStreamSynchronize(st));   // dmap is freed on return
    ++launches;
}

// y[row, dst_col] = sign * x[row, src_col] for every column of a block: the
// down-spin creation / annihilation operators, which act inside a row.  Map
// entry per destination down state (src_col << 1) | neg, or -1 for zero; every
// entry also takes (-1)^{n_up} (neg_all), the up orbitals the operator passes in
// the Jordan-Wigner order.
template <typename VS, typename VD>
__global__ void __launch_bounds__(256) k_colmap(const VS* __restrict__ x, VD* __restrict__ y,
                                                const int32_t* __restrict__ map, int64_t Dup, int64_t Dsrc,
                                                int64_t Ddst, int neg_all, int64_t ld_x, int64_t ld_y) {
    const int64_t n = Dup * Ddst;
    const VS* __restrict__ xc = x + int64_t(blockIdx.y) * ld_x;
    VD* __restrict__ yc = y + int64_t(blockIdx.y) * ld_y;
    for (int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; s < n; s += int64_t(gridDim.x) * blockDim.x) {
        const int64_t u = s / Ddst, d = s - u * Ddst;
        const int32_t m = __ldg(map + d);
        VD out = vzero(VD{});
        if (m >= 0) {
            const VS v = xc[u * Dsrc + (m >> 1)];
            if constexpr (is_cplx_v<VS>) {
                out = mk(scalar_t<VD>(v.x), scalar_t<VD>(v.y));
            } else {
                out = mk(scalar_t<VD>(v), scalar_t<VD>(0));
            }
            if ((m & 1) ^ neg_all) out = vsub(vzero(VD{}), out);
        }
        yc[s] = out;
    }
}

template <typename VS, typename VD>
static void launch_colmap(const VS* x, VD* y, const std::vector<int32_t>& map, int64_t Dup, int64_t Dsrc, int neg_all,
                          int64_t ld_x, int64_t ld_y, int nvec, cudaStream_t st, int64_t& launches) {
    DevBuf<int32_t> dmap(map.size());
    dmap.upload(map.data(), map.size(), st);
    const int64_t Ddst = int64_t(map.size());
    const int64_t n = Dup * Ddst;
    {
        ProfScope ps("sector_map", st, double(nvec) * n * (sizeof(VS) + sizeof(VD)), 0);
        k_colmap<VS, VD><<<dim3(grid_for(n, 256, 8), nvec), 256, 0, st>>>(x, y, dmap.p, Dup, Dsrc, Ddst, neg_all, ld_x,
                                                                           ld_y);
    }
    MSB_LAUNCH_CHECK();
    MSB_CUDA(cudaStreamSynchronize(st));   // dmap is freed on return
    ++launches;
}

// y = c^dag_{j,spin} x (create) or c_{j,spin} x for nvec vectors of the (nu, nd) sector
// (vector strides ld_x, ld_y): up spin maps rows, down spin maps the columns of a row.
template <typename VS, typename VD>
static void launch_sector_op(const VS* x, VD* y, int L, int nu, int nd, int j, int spin, bool create, int64_t ld_x,
                             int64_t ld_y, int nvec, cudaStream_t st, int64_t& launches) {
    if (spin == 0) {
        MSB_REQUIRE(create ? nu + 1 <= L : nu >= 1, "no up electron to create / annihilate");
        auto map = create ? cdag_rowmap(L, nu, j) : c_rowmap(L, nu - 1, j);
        const int64_t Ddn = int64_t(sector_states(L, nd).size());
        launch_rowmap(x, y, map, Ddn, ld_x, ld_y, nvec, st, launches);
    } else {
        MSB_REQUIRE(create ? nd + 1 <= L : nd >= 1, "no down electron to create / annihilate");
        auto map = create ? cdag_rowmap(L, nd, j) : c_rowmap(L, nd - 1, j);
        const int64_t Dup = int64_t(sector_states(L, nu).size()), Dsrc = int64_t(sector_states(L, nd).size());
        launch_colmap(x, y, map, Dup, Dsrc, nu & 1, ld_x, ld_y, nvec, st, launches);
    }
}

static void apply_sector_map(const msb_model& m, int site, bool create, const void* x, void* y, int nvec,
                             msb_precision prec, cudaStream_t st) {
    validate_model(m);
    MSB_REQUIRE(site >= 0 && site < m.L, "site must be in 0..L-1");
    MSB_REQUIRE(m.n_up + 1 <= m.L, "need n_up + 1 <= L");
    MSB_REQUIRE(x && y && nvec >= 1 && nvec <= 65535, "invalid vectors");
    const int64_t Ddn = int64_t(sector_states(m.L, m.n_dn).size());
    const int64_t Dlo = int64_t(sector_states(m.L, m.n_up).size()) * Ddn;
    const int64_t Dhi = int64_t(sector_states(m.L, m.n_up + 1).size()) * Ddn;
    auto map = create ? cdag_rowmap(m.L, m.n_up, site) : c_rowmap(m.L, m.n_up, site);
    const int64_t ldx = create ? Dlo : Dhi, ldy = create ? Dhi : Dlo;
    int64_t launches = 0;
    if (prec == MSB_FP64)
        launch_rowmap((const double2*)x, (double2*)y, map, Ddn, ldx, ldy, nvec, st, launches);
    else
        launch_rowmap((const float2*)x, (float2*)y, map, Ddn, ldx, ldy, nvec, st, launches);
}

// ---------------------------------------------------------------------------
// The map
// ---------------------------------------------------------------------------
// Steps 3-5 of the map for one core site (m.core_site): E = O2|G>, the
// multi-shift solve on H' of that site, and phi_k = O1 Psi_k written to Phi
// (n_in vectors of the final sector, precision of prm).  Returns the solve status.
// O2 = c^dag_{j,o2_spin}, O1 = c_{j,o1_spin}.  With an up-spin O1 only the rows of
// the intermediate sector that O1 reads (site j up-occupied) are carried per shift,
// since the per-shift update is elementwise; a down-spin O1 acts inside every row.
static msb_status solve_site(msb_op* opHp, const msb_op* opH, const msb_op* opHf, const msb_model& m,
                             const msb_map_params& prm, const double* G, double E_G, const double* w_in, int n_in,
                             char* Phi, msb_solve_info& info, cudaStream_t st, int64_t& launches) {
    const int64_t D = opH->dim, Dp = opHp->dim, Df = opHf->dim;
    const int j = m.core_site;
    int nu_i = 0, nd_i = 0;
    model_sector(m, 1, nu_i, nd_i);
    const int64_t Ddn_i = opHp->hub.Ddn;
    const size_t csz = prm.precision == MSB_FP64 ? sizeof(double2) : sizeof(float2);
    DevBuf<char> Ebuf(size_t(Dp) * csz);
    if (prm.precision == MSB_FP64)
        launch_sector_op(G, (double2*)Ebuf.p, m.L, m.n_up, m.n_dn, j, m.o2_spin, true, D, Dp, 1, st, launches);
    else
        launch_sector_op(G, (float2*)Ebuf.p, m.L, m.n_up, m.n_dn, j, m.o2_spin, true, D, Dp, 1, st, launches);
    // rows of the intermediate sector that an up-spin O1 reads (site j up-occupied)
    const auto up_hi = sector_states(m.L, nu_i);
    std::vector<int32_t> rows;
    std::vector<int32_t> pos(up_hi.size(), -1);
    if (m.o1_spin == 0)
        for (size_t r = 0; r < up_hi.size(); ++r)
            if ((up_hi[r] >> j) & 1u) { pos[r] = int32_t(rows.size()); rows.push_back(int32_t(r)); }
    DevBuf<int32_t> drows(rows.size());
    if (!rows.empty()) drows.upload(rows.data(), rows.size(), st);
    const int64_t n_out = m.o1_spin == 0 ? int64_t(rows.size()) * Ddn_i : Dp;
    // seed and shifts
    int s0 = prm.seed_index;
    if (s0 < 0) {
        s0 = 0;
        for (int k = 1; k < n_in; ++k) if (std::fabs(w_in[k]) < std::fabs(w_in[s0])) s0 = k;
    }
    MSB_REQUIRE(s0 < n_in, "seed_index out of range");
    SolveProblem pr;
    pr.n = Dp;
    pr.ns = n_in;
    pr.b = Ebuf.p;
    pr.n_out = n_out;
    pr.rows = m.o1_spin == 0 ? drows.p : nullptr;
    pr.rowlen = Ddn_i;
    pr.c0 = make_double2(-E_G - w_in[s0], -prm.Gamma);
    pr.tol = prm.solve_tol;
    pr.maxit = prm.maxit;
    pr.block = pick_block(prm.block, prm.precision, pr.n, pr.ns);
    pr.prec = prm.precision;
    pr.shifts.resize(n_in);
    for (int k = 0; k < n_in; ++k) pr.shifts[k] = make_double2(w_in[k] - w_in[s0], 0.0);
    DevBuf<char> Xsub(size_t(n_in) * n_out * csz);
    pr.x = Xsub.p;
    SolveResult sr;
    multishift_solve(opHp, pr, sr, st);
    MSB_CUDA(cudaStreamSynchronize(st));
    launches += sr.launches;
    info.iterations = std::max(info.iterations, sr.iterations);
    info.n_converged += sr.n_converged;
    info.flushes += sr.flushes;
    info.seed_residual = std::max(info.seed_residual, sr.seed_residual);
    for (double r : sr.resid) info.max_shift_residual = std::max(info.max_shift_residual, r);
    info.matvecs += sr.iterations;
    if (sr.status != MSB_OK && sr.status != MSB_EMAXITER) fail(sr.status, "multi-shift solve failed");
    Ebuf.release();
    // phi_k = O1 Psi_k
    if (m.o1_spin == 0) {
        std::vector<int32_t> omap(size_t(Df / Ddn_i), -1);
        const auto up_lo = sector_states(m.L, nu_i - 1);
        MSB_REQUIRE(int64_t(up_lo.size()) * Ddn_i == Df, "final sector size mismatch");
        auto rhi = rank_table(up_hi, m.L);
        for (size_t r = 0; r < up_lo.size(); ++r) {
            const uint32_t u = up_lo[r];
            if ((u >> j) & 1u) continue;
            const int32_t src = pos[rhi[u | (1u << j)]];
            omap[r] = (src << 1) | jw_sign_below(u, j);
        }
        if (prm.precision == MSB_FP64)
            launch_rowmap((const double2*)Xsub.p, (double2*)Phi, omap, Ddn_i, n_out, Df, n_in, st, launches);
        else
            launch_rowmap((const float2*)Xsub.p, (float2*)Phi, omap, Ddn_i, n_out, Df, n_in, st, launches);
    } else {
        if (prm.precision == MSB_FP64)
            launch_sector_op((const double2*)Xsub.p, (double2*)Phi, m.L, nu_i, nd_i, j, 1, false, Dp, Df, n_in, st,
                             launches);
        else
            launch_sector_op((const float2*)Xsub.p, (float2*)Phi, m.L, nu_i, nd_i, j, 1, false, Dp, Df, n_in, st,
                             launches);
    }
    return sr.status;
}

void rixs_map_core(msb_op* opH, msb_op* opHp, const msb_model& m, const msb_map_params& prm, const double* G_in,
                   double E_G_in, const double* w_in, int n_in, const double* w, int n_w, double* I_out, bool I_dev,
                   msb_solve_info& info, cudaStream_t st, int64_t launches_so_far);

void rixs_map(const msb_model& m, const msb_map_params& prm, const double* G_in, double E_G_in, const double* w_in,
              int n_in, const double* w, int n_w, double* I_out, msb_solve_info& info, cudaStream_t st) {
    validate_model(m);
    std::unique_ptr<msb_op> opH, opHp;
    {
        msb_op* a = nullptr;
        msb_status s1 = msb_op_create_hubbard(&m, 0, &a);
        if (s1 != MSB_OK) fail(s1, msb_last_error());
        opH.reset(a);
        s1 = msb_op_create_hubbard(&m, 1, &a);
        if (s1 != MSB_OK) fail(s1, msb_last_error());
        opHp.reset(a);
    }
    rixs_map_core(opH.get(), opHp.get(), m, prm, G_in, E_G_in, w_in, n_in, w, n_w, I_out, false, info, st, 0);
}

void rixs_map_core(msb_op* opH_, msb_op* opHp_, const msb_model& m, const msb_map_params& prm, const double* G_in,
                   double E_G_in, const double* w_in, int n_in, const double* w, int n_w, double* I_out, bool I_dev,
                   msb_solve_info& info, cudaStream_t st, int64_t launches_so_far) {
    validate_model(m);
    MSB_REQUIRE(m.flux == 0.0, "the map needs a real H (no flux): the dual solver takes complex H");
    MSB_REQUIRE(n_in >= 1 && n_in <= kMaxShifts, "n_in must be in 1..4096");
    MSB_REQUIRE(n_w >= 1, "n_w must be >= 1");
    MSB_REQUIRE(w_in && w && I_out, "NULL argument");
    MSB_REQUIRE(prm.Gamma > 0 && prm.eta > 0, "Gamma and eta must be > 0");
    MSB_REQUIRE(prm.precision == MSB_FP64 || prm.precision == MSB_FP32_MIXED, "unknown precision");
    const auto t_start = std::chrono::steady_clock::now();
    auto secs = [](std::chrono::steady_clock::time_point a) {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - a).count();
    };
    int64_t launches = launches_so_far;
    struct { msb_op* get() const { return p; } msb_op* operator->() const { return p; } msb_op* p; } opH{opH_},
        opHp{opHp_};
    const int64_t D = opH->dim;

    // ground state
    auto t0 = std::chrono::steady_clock::now();
    DevBuf<double> gbuf;
    const double* G = G_in;
    double E_G = E_G_in;
    if (!G) {
        gbuf.alloc(D);
        GroundResult gr;
        ground_state(opH.get(), prm.gs_tol, prm.gs_maxit, nullptr, gbuf.p, gr, st);
        if (gr.status != MSB_OK) fail(gr.status, "ground state: tolerance not reached");
        G = gbuf.p;
        E_G = gr.E;
        info.gs_residual = gr.residual;
        info.matvecs += gr.matvecs;
        launches += gr.launches;
    }
    info.E_G = E_G;
    info.seconds_ground_state = secs(t0);

    // the final sector: the ground sector in the spin-conserving channel
    std::unique_ptr<msb_op> opHf_own;
    msb_op* opHf = opH.get();
    if (m.o1_spin != m.o2_spin) {
        msb_op* a = nullptr;
        const msb_status s1 = msb_op_create_hubbard(&m, 2, &a);
        if (s1 != MSB_OK) fail(s1, msb_last_error());
        opHf_own.reset(a);
        opHf = a;
    }
    // E = O2 |G>, the multi-shift solve, phi = O1 Psi
    t0 = std::chrono::steady_clock::now();
    const size_t csz = prm.precision == MSB_FP64 ? sizeof(double2) : sizeof(float2);
    DevBuf<char> Phi(size_t(n_in) * opHf->dim * csz);
    const msb_status sst =
        solve_site(opHp.get(), opH.get(), opHf, m, prm, G, E_G, w_in, n_in, Phi.p, info, st, launches);
    info.seconds_solve = secs(t0);

    // second step, on the final sector's H
    t0 = std::chrono::steady_clock::now();
    CFResult cr;
    continued_fraction(opHf, Phi.p, n_in, E_G, w, n_w, prm.eta, prm.cf_tol, prm.cf_check, prm.cf_maxdepth,
                       prm.precision, I_out, cr, st, I_dev);
    launches += cr.launches;
    info.matvecs += cr.matvecs;
    int dmax = 0, dmin = 1 << 30;
    for (int d : cr.depth) { dmax = std::max(dmax, d); dmin = std::min(dmin, d); }
    info.cf_depth_max = dmax;
    info.cf_depth_min = dmin;
    info.seconds_second_step = secs(t0);
    info.seconds_total = secs(t_start);
    info.kernel_launches = launches;
    if (sst == MSB_EMAXITER) fail(MSB_EMAXITER, "some incident energies did not converge (map written)");
}

}  // namespace msb

extern "C" msb_status msb_apply_cdag_up(const msb_model* model, int site, const void* x, void* y, int nvec,
                                        msb_precision prec, void* stream) {
    return msb::guard("msb_apply_cdag_up", [&] {
        msb::require_device();
        MSB_REQUIRE(model != nullptr, "model is NULL");
        msb::apply_sector_map(*model, site, true, x, y, nvec, prec, (cudaStream_t)stream);
    });
}

extern "C" msb_status msb_apply_c_up(const msb_model* model, int site, const void* x, void* y, int nvec,
                                     msb_precision prec, void* stream) {
    return msb::guard("msb_apply_c_up", [&] {
        msb::require_device();
        MSB_REQUIRE(model != nullptr, "model is NULL");
        msb::apply_sector_map(*model, site, false, x, y, nvec, prec, (cudaStream_t)stream);
    });
}

namespace msb {

// Maps of several core sites of one model (one right-hand side O2 = c^dag_{j,up}
// per site): one ground state, one solve per site on its own H', then one
// continued fraction over all sites' columns, since H is the same for all.
// phi_q = sum_j exp(i q site_j) phi_j for every momentum q, incident energy and
// element: out[q][r] = sum_j ph[q][j] phi[j][r], r < per_site (= n_in * D).
template <typename C>
__global__ void __launch_bounds__(256) k_qsum(const C* __restrict__ phi, int n_sites, int64_t per_site,
                                              const double2* __restrict__ ph, int n_q, C* __restrict__ out) {
    using S = scalar_t<C>;
    const int64_t n = int64_t(n_q) * per_site;
    for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < n; e += int64_t(gridDim.x) * blockDim.x) {
        const int q = int(e / per_site);
        const int64_t r = e - int64_t(q) * per_site;
        S ax = S(0), ay = S(0);
        for (int j = 0; j < n_sites; ++j) {
            const double2 p = ph[int64_t(q) * n_sites + j];
            const C v = phi[int64_t(j) * per_site + r];
            ax += S(p.x) * v.x - S(p.y) * v.y;
            ay += S(p.x) * v.y + S(p.y) * v.x;
        }
        out[e] = mk(ax, ay);
    }
}

// Steps 3-5 for several core sites j of one model in ONE multi-shift solve: the
// block-diagonal operator A = (+)_j (H'_j - E_G) (one block per core site, each
// with its own core hole) and the concatenated right-hand side (O2_j |G>)_j.  The
// Krylov space of A keeps the blocks apart, so one recurrence (Alg. 1) solves
// every site at every incident energy, and each launch of the solve covers all
// sites.  Per-shift vectors carry only the rows each site's O1 reads.  The joint
// residual bound tol * min_j ||b_j|| / ||b|| meets every site's own bound.
// Phi: n_sites x n_in vectors of the ground sector (site slowest).
static msb_status solve_sites_joint(const msb_op* opH, const msb_model& m, const msb_map_params& prm,
                                    const int* sites, int n_sites, const double* G, double E_G, const double* w_in,
                                    int n_in, char* Phi, msb_solve_info& info, cudaStream_t st, int64_t& launches) {
    MSB_REQUIRE(n_sites >= 1 && n_sites <= kMaxParts, "need 1..16 core sites");
    const int64_t D = opH->dim, Ddn = opH->hub.Ddn;
    const size_t csz = prm.precision == MSB_FP64 ? sizeof(double2) : sizeof(float2);
    std::vector<std::unique_ptr<msb_op>> opHp(n_sites);
    for (int i = 0; i < n_sites; ++i) {
        msb_model mj = m;
        mj.core_site = sites[i];
        msb_op* b = nullptr;
        const msb_status s1 = msb_op_create_hubbard(&mj, 1, &b);
        if (s1 != MSB_OK) fail(s1, msb_last_error());
        opHp[i].reset(b);
    }
    const int64_t Dp = opHp[0]->dim;
    const int64_t n = int64_t(n_sites) * Dp;
    // right-hand side (O2_j |G>)_j; every block has norm ||c_{j,up}^dag G||
    DevBuf<char> Ebuf(size_t(n) * csz);
    std::vector<double> hg(D);
    MSB_CUDA(cudaMemcpyAsync(hg.data(), G, D * sizeof(double), cudaMemcpyDeviceToHost, st));
    MSB_CUDA(cudaStreamSynchronize(st));
    double bmin = 0, b2 = 0;
    // rows carried per shift: block i, intermediate up-rows with site j up-occupied
    const auto up_hi = sector_states(m.L, m.n_up + 1);
    const int64_t Dup_hi = int64_t(up_hi.size());
    std::vector<int32_t> rows;
    std::vector<std::vector<int32_t>> pos(n_sites, std::vector<int32_t>(up_hi.size(), -1));
    for (int i = 0; i < n_sites; ++i) {
        const int j = sites[i];
        auto map = cdag_rowmap(m.L, m.n_up, j);
        char* dst = Ebuf.p + size_t(i) * Dp * csz;
        if (prm.precision == MSB_FP64)
            launch_rowmap(G, (double2*)dst, map, Ddn, D, Dp, 1, st, launches);
        else
            launch_rowmap(G, (float2*)dst, map, Ddn, D, Dp, 1, st, launches);
        double nb = 0;
        for (size_t r = 0; r < map.size(); ++r) {
            if (map[r] < 0) continue;
            const double* gp = hg.data() + int64_t(map[r] >> 1) * Ddn;
            for (int64_t d = 0; d < Ddn; ++d) nb += gp[d] * gp[d];
        }
        MSB_REQUIRE(nb > 0, "O2 annihilates the ground state (no intermediate state)");
        bmin = i == 0 ? std::sqrt(nb) : std::min(bmin, std::sqrt(nb));
        b2 += nb;
        for (int64_t r = 0; r < Dup_hi; ++r)
            if ((up_hi[r] >> j) & 1u) {
                pos[i][r] = int32_t(rows.size());
                rows.push_back(int32_t(int64_t(i) * Dup_hi + r));
            }
    }
    DevBuf<int32_t> drows(rows.size());
    drows.upload(rows.data(), rows.size(), st);
    const int64_t n_out = int64_t(rows.size()) * Ddn;
    std::vector<const msb_op*> parts(n_sites);
    std::vector<double> shifts(n_sites, -E_G);
    for (int i = 0; i < n_sites; ++i) parts[i] = opHp[i].get();
    std::unique_ptr<msb_op> A;
    {
        msb_op* a = nullptr;
        const msb_status s1 = msb_op_create_direct_sum(parts.data(), shifts.data(), n_sites, &a);
        if (s1 != MSB_OK) fail(s1, msb_last_error());
        A.reset(a);
    }
    int s0 = prm.seed_index;
    if (s0 < 0) {
        s0 = 0;
        for (int k = 1; k < n_in; ++k) if (std::fabs(w_in[k]) < std::fabs(w_in[s0])) s0 = k;
    }
    MSB_REQUIRE(s0 < n_in, "seed_index out of range");
    SolveProblem pr;
    pr.n = n;
    pr.ns = n_in;
    pr.b = Ebuf.p;
    pr.n_out = n_out;
    pr.rows = drows.p;
    pr.rowlen = Ddn;
    pr.c0 = make_double2(-w_in[s0], -prm.Gamma);
    pr.tol = prm.solve_tol * bmin / std::sqrt(b2);
    pr.maxit = prm.maxit;
    pr.block = pick_block(prm.block, prm.precision, pr.n, pr.ns);
    pr.prec = prm.precision;
    pr.shifts.resize(n_in);
    for (int k = 0; k < n_in; ++k) pr.shifts[k] = make_double2(w_in[k] - w_in[s0], 0.0);
    DevBuf<char> X(size_t(n_in) * n_out * csz);
    pr.x = X.p;
    SolveResult sr;
    multishift_solve(A.get(), pr, sr, st);
    MSB_CUDA(cudaStreamSynchronize(st));
    launches += sr.launches;
    info.iterations = std::max(info.iterations, sr.iterations);
    info.n_converged += sr.n_converged;
    info.flushes += sr.flushes;
    info.seed_residual = std::max(info.seed_residual, sr.seed_residual);
    for (double r : sr.resid) info.max_shift_residual = std::max(info.max_shift_residual, r);
    info.matvecs += sr.iterations;
    if (sr.status != MSB_OK && sr.status != MSB_EMAXITER) fail(sr.status, "multi-shift solve failed");
    Ebuf.release();
    // phi_{j,k} = O1_j Psi_{j,k} from the carried rows
    const auto up_lo = sector_states(m.L, m.n_up);
    auto rhi = rank_table(up_hi, m.L);
    for (int i = 0; i < n_sites; ++i) {
        const int j = sites[i];
        std::vector<int32_t> omap(opH->hub.Dup, -1);
        for (size_t r = 0; r < up_lo.size(); ++r) {
            const uint32_t u = up_lo[r];
            if ((u >> j) & 1u) continue;
            const int32_t src = pos[i][rhi[u | (1u << j)]];
            omap[r] = (src << 1) | jw_sign_below(u, j);
        }
        char* dst = Phi + size_t(i) * n_in * D * csz;
        if (prm.precision == MSB_FP64)
            launch_rowmap((const double2*)X.p, (double2*)dst, omap, Ddn, n_out, D, n_in, st, launches);
        else
            launch_rowmap((const float2*)X.p, (float2*)dst, omap, Ddn, n_out, D, n_in, st, launches);
    }
    return sr.status;
}

// Maps of several core sites (n_q = 0: one map per site), or their coherent sums
// over the sites with momentum phases (n_q > 0: one map per q, Sec. III).
static void rixs_map_sites_impl(const msb_model& m, const msb_map_params& prm, const int* sites, int n_sites,
                                const double* w_in, int n_in, const double* w, int n_w, double* I_out,
                                msb_solve_info& info, cudaStream_t st, const double* qs = nullptr,
                                int n_q = 0) {
    validate_model(m);
    MSB_REQUIRE(m.o2_spin == 0 && m.o1_spin == 0, "the site batch supports the up-spin channel");
    MSB_REQUIRE(m.flux == 0.0, "the map needs a real H (no flux)");
    MSB_REQUIRE(sites != nullptr && n_sites >= 1, "need at least one site");
    MSB_REQUIRE(n_in >= 1 && n_in <= kMaxShifts && int64_t(n_sites) * n_in <= 65535,
                "n_sites * n_in must be at most 65535 (and n_in at most 4096)");
    MSB_REQUIRE(m.n_up + 1 <= m.L, "the intermediate sector needs n_up + 1 <= L");
    MSB_REQUIRE(w_in && w && I_out && n_w >= 1, "NULL argument");
    MSB_REQUIRE(prm.Gamma > 0 && prm.eta > 0, "Gamma and eta must be > 0");
    for (int i = 0; i < n_sites; ++i) MSB_REQUIRE(sites[i] >= 0 && sites[i] < m.L, "site out of range");
    const auto t_start = std::chrono::steady_clock::now();
    auto secs = [](std::chrono::steady_clock::time_point a) {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - a).count();
    };
    int64_t launches = 0;
    msb_op* a = nullptr;
    msb_status s1 = msb_op_create_hubbard(&m, 0, &a);
    if (s1 != MSB_OK) fail(s1, msb_last_error());
    std::unique_ptr<msb_op> opH(a);
    const int64_t D = opH->dim;
    auto t0 = std::chrono::steady_clock::now();
    DevBuf<double> g(D);
    GroundResult gr;
    ground_state(opH.get(), prm.gs_tol, prm.gs_maxit, nullptr, g.p, gr, st);
    if (gr.status != MSB_OK) fail(gr.status, "ground state: tolerance not reached");
    info.E_G = gr.E;
    info.gs_residual = gr.residual;
    info.matvecs += gr.matvecs;
    launches += gr.launches;
    info.seconds_ground_state = secs(t0);
    t0 = std::chrono::steady_clock::now();
    const size_t csz = prm.precision == MSB_FP64 ? sizeof(double2) : sizeof(float2);
    DevBuf<char> Phi(size_t(n_sites) * n_in * D * csz);
    const msb_status sst = solve_sites_joint(opH.get(), m, prm, sites, n_sites, g.p, gr.E, w_in, n_in, Phi.p, info,
                                             st, launches);
    const bool maxit_hit = sst == MSB_EMAXITER;
    const void* cf_in = Phi.p;
    int n_cols = n_sites * n_in;
    DevBuf<char> Phiq;
    if (n_q > 0) {
        std::vector<double2> ph(size_t(n_q) * n_sites);
        for (int q = 0; q < n_q; ++q)
            for (int j = 0; j < n_sites; ++j)
                ph[size_t(q) * n_sites + j] = make_double2(std::cos(qs[q] * sites[j]), std::sin(qs[q] * sites[j]));
        DevBuf<double2> dph(ph.size());
        dph.upload(ph.data(), ph.size(), st);
        const int64_t per_site = int64_t(n_in) * D;
        Phiq.alloc(size_t(n_q) * per_site * csz);
        const int g = grid_for(int64_t(n_q) * per_site, 256, 8);
        {
            ProfScope ps("sector_map", st, double(n_q) * per_site * csz * (n_sites + 1), 8.0 * n_q * per_site * n_sites);
            if (prm.precision == MSB_FP64)
                k_qsum<double2><<<g, 256, 0, st>>>((const double2*)Phi.p, n_sites, per_site, dph.p, n_q,
                                                   (double2*)Phiq.p);
            else
                k_qsum<float2><<<g, 256, 0, st>>>((const float2*)Phi.p, n_sites, per_site, dph.p, n_q,
                                                  (float2*)Phiq.p);
        }
        MSB_LAUNCH_CHECK();
        MSB_CUDA(cudaStreamSynchronize(st));
        ++launches;
        Phi.release();
        cf_in = Phiq.p;
        n_cols = n_q * n_in;
    }
    info.seconds_solve = secs(t0);
    t0 = std::chrono::steady_clock::now();
    CFResult cr;
    continued_fraction(opH.get(), cf_in, n_cols, gr.E, w, n_w, prm.eta, prm.cf_tol, prm.cf_check,
                       prm.cf_maxdepth, prm.precision, I_out, cr, st, false);
    launches += cr.launches;
    info.matvecs += cr.matvecs;
    int dmax = 0, dmin = 1 << 30;
    for (int d : cr.depth) { dmax = std::max(dmax, d); dmin = std::min(dmin, d); }
    info.cf_depth_max = dmax;
    info.cf_depth_min = dmin;
    info.seconds_second_step = secs(t0);
    info.seconds_total = secs(t_start);
    info.kernel_launches = launches;
    if (maxit_hit) fail(MSB_EMAXITER, "some incident energies did not converge (maps written)");
}

// Maps of several independent clusters (uneven sizes) in one solve and one
// continued fraction.  The direct sum A = (+)_c (H'_c - E_G,c) makes the seed
// system (A - w_seed - i Gamma) carry each cluster's own energy origin while the
// shifts w_in - w_seed stay common, so one Krylov recurrence (Alg. 1) on the
// concatenated right-hand side (O2 |G_c>)_c solves every cluster and every
// incident energy: the block-diagonal A keeps the clusters' components apart.
// ||r_c|| <= ||r||, so the joint bound tol * min_c ||b_c|| meets each cluster's.
static void rixs_map_clusters_impl(const msb_model* models, int nc, const msb_map_params& prm, const double* w_in,
                                   int n_in, const double* w, int n_w, double* I_out, double* E_out,
                                   msb_solve_info& info, cudaStream_t st) {
    MSB_REQUIRE(models != nullptr && nc >= 1 && nc <= kMaxParts, "need 1..16 clusters");
    MSB_REQUIRE(n_in >= 1 && n_in <= kMaxShifts && int64_t(nc) * n_in <= 65535,
                "n_clusters * n_in must be at most 65535 (and n_in at most 4096)");
    MSB_REQUIRE(w_in && w && I_out && n_w >= 1, "NULL argument");
    MSB_REQUIRE(prm.Gamma > 0 && prm.eta > 0, "Gamma and eta must be > 0");
    MSB_REQUIRE(prm.precision == MSB_FP64 || prm.precision == MSB_FP32_MIXED, "unknown precision");
    for (int c = 0; c < nc; ++c) {
        validate_model(models[c]);
        MSB_REQUIRE(models[c].o2_spin == 0 && models[c].o1_spin == 0, "the cluster batch supports the up-spin channel");
        MSB_REQUIRE(models[c].flux == 0.0, "the map needs a real H (no flux)");
        MSB_REQUIRE(models[c].n_up + 1 <= models[c].L, "the intermediate sector needs n_up + 1 <= L");
        MSB_REQUIRE(models[c].core_site >= 0 && models[c].core_site < models[c].L, "core_site out of range");
    }
    const auto t_start = std::chrono::steady_clock::now();
    auto secs = [](std::chrono::steady_clock::time_point a) {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - a).count();
    };
    int64_t launches = 0;
    std::vector<std::unique_ptr<msb_op>> opH(nc), opHp(nc);
    for (int c = 0; c < nc; ++c) {
        msb_op* a = nullptr;
        msb_status s1 = msb_op_create_hubbard(&models[c], 0, &a);
        if (s1 != MSB_OK) fail(s1, msb_last_error());
        opH[c].reset(a);
        s1 = msb_op_create_hubbard(&models[c], 1, &a);
        if (s1 != MSB_OK) fail(s1, msb_last_error());
        opHp[c].reset(a);
    }
    // ground states, one per cluster
    auto t0 = std::chrono::steady_clock::now();
    std::vector<DevBuf<double>> G(nc);
    std::vector<double> EG(nc);
    for (int c = 0; c < nc; ++c) {
        G[c].alloc(opH[c]->dim);
        GroundResult gr;
        ground_state(opH[c].get(), prm.gs_tol, prm.gs_maxit, nullptr, G[c].p, gr, st);
        if (gr.status != MSB_OK) fail(gr.status, "ground state: tolerance not reached");
        EG[c] = gr.E;
        info.gs_residual = std::max(info.gs_residual, gr.residual);
        info.matvecs += gr.matvecs;
        launches += gr.launches;
        if (E_out) E_out[c] = gr.E;
    }
    info.E_G = EG[0];
    info.seconds_ground_state = secs(t0);

    // concatenated right-hand side (O2 |G_c>)_c and its per-cluster norms
    t0 = std::chrono::steady_clock::now();
    const size_t csz = prm.precision == MSB_FP64 ? sizeof(double2) : sizeof(float2);
    std::vector<int64_t> offp(nc + 1, 0);
    for (int c = 0; c < nc; ++c) offp[c + 1] = offp[c] + opHp[c]->dim;
    const int64_t n = offp[nc];
    DevBuf<char> Ebuf(size_t(n) * csz);
    double bmin = 0, b2 = 0;
    for (int c = 0; c < nc; ++c) {
        const msb_model& m = models[c];
        const int64_t D = opH[c]->dim, Ddn = opH[c]->hub.Ddn;
        auto map = cdag_rowmap(m.L, m.n_up, m.core_site);
        char* dst = Ebuf.p + size_t(offp[c]) * csz;
        if (prm.precision == MSB_FP64)
            launch_rowmap(G[c].p, (double2*)dst, map, Ddn, D, opHp[c]->dim, 1, st, launches);
        else
            launch_rowmap(G[c].p, (float2*)dst, map, Ddn, D, opHp[c]->dim, 1, st, launches);
        std::vector<double> hg(D);
        MSB_CUDA(cudaMemcpyAsync(hg.data(), G[c].p, D * sizeof(double), cudaMemcpyDeviceToHost, st));
        MSB_CUDA(cudaStreamSynchronize(st));
        double nb = 0;
        for (size_t r = 0; r < map.size(); ++r) {
            if (map[r] < 0) continue;
            const double* g = hg.data() + int64_t(map[r] >> 1) * Ddn;
            for (int64_t d = 0; d < Ddn; ++d) nb += g[d] * g[d];
        }
        MSB_REQUIRE(nb > 0, "O2 annihilates the ground state of a cluster (no intermediate state)");
        bmin = c == 0 ? std::sqrt(nb) : std::min(bmin, std::sqrt(nb));
        b2 += nb;
    }
    // the direct sum and the joint solve
    std::vector<const msb_op*> parts(nc);
    std::vector<double> shifts(nc);
    for (int c = 0; c < nc; ++c) { parts[c] = opHp[c].get(); shifts[c] = -EG[c]; }
    std::unique_ptr<msb_op> A;
    {
        msb_op* a = nullptr;
        const msb_status s1 = msb_op_create_direct_sum(parts.data(), shifts.data(), nc, &a);
        if (s1 != MSB_OK) fail(s1, msb_last_error());
        A.reset(a);
    }
    int s0 = prm.seed_index;
    if (s0 < 0) {
        s0 = 0;
        for (int k = 1; k < n_in; ++k) if (std::fabs(w_in[k]) < std::fabs(w_in[s0])) s0 = k;
    }
    MSB_REQUIRE(s0 < n_in, "seed_index out of range");
    SolveProblem pr;
    pr.n = n;
    pr.ns = n_in;
    pr.b = Ebuf.p;
    pr.n_out = n;
    pr.c0 = make_double2(-w_in[s0], -prm.Gamma);
    pr.tol = prm.solve_tol * bmin / std::sqrt(b2);
    pr.maxit = prm.maxit;
    pr.block = pick_block(prm.block, prm.precision, pr.n, pr.ns);
    pr.prec = prm.precision;
    pr.shifts.resize(n_in);
    for (int k = 0; k < n_in; ++k) pr.shifts[k] = make_double2(w_in[k] - w_in[s0], 0.0);
    DevBuf<char> X(size_t(n_in) * n * csz);
    pr.x = X.p;
    SolveResult sr;
    multishift_solve(A.get(), pr, sr, st);
    MSB_CUDA(cudaStreamSynchronize(st));
    launches += sr.launches;
    info.iterations = sr.iterations;
    info.n_converged = sr.n_converged;
    info.flushes = sr.flushes;
    info.seed_residual = sr.seed_residual;
    for (double r : sr.resid) info.max_shift_residual = std::max(info.max_shift_residual, r);
    info.matvecs += sr.iterations;
    if (sr.status != MSB_OK && sr.status != MSB_EMAXITER) fail(sr.status, "multi-shift solve failed");
    Ebuf.release();
    // phi_{c,k} = O1 Psi_{c,k}, column c * n_in + k, stride ldphi
    int64_t ldphi = 0;
    for (int c = 0; c < nc; ++c) ldphi = std::max(ldphi, opH[c]->dim);
    DevBuf<char> Phi(size_t(nc) * n_in * ldphi * csz);
    for (int c = 0; c < nc; ++c) {
        const msb_model& m = models[c];
        auto omap = c_rowmap(m.L, m.n_up, m.core_site);
        const int64_t Ddn = opH[c]->hub.Ddn;
        const char* src = X.p + size_t(offp[c]) * csz;
        char* dst = Phi.p + size_t(c) * n_in * ldphi * csz;
        if (prm.precision == MSB_FP64)
            launch_rowmap((const double2*)src, (double2*)dst, omap, Ddn, n, ldphi, n_in, st, launches);
        else
            launch_rowmap((const float2*)src, (float2*)dst, omap, Ddn, n, ldphi, n_in, st, launches);
    }
    X.release();
    info.seconds_solve = secs(t0);
    // one continued fraction over every cluster's columns
    t0 = std::chrono::steady_clock::now();
    CFColumns P;
    P.phi = Phi.p;
    P.ldphi = ldphi;
    P.nv = nc * n_in;
    for (int c = 0; c < nc; ++c) P.ops.push_back(opH[c].get());
    for (int c = 0; c < nc; ++c)
        for (int k = 0; k < n_in; ++k) {
            P.q.push_back(c);
            P.E0.push_back(EG[c]);
        }
    CFResult cr;
    continued_fraction_columns(P, w, n_w, prm.eta, prm.cf_tol, prm.cf_check, prm.cf_maxdepth, prm.precision, I_out,
                               cr, st);
    launches += cr.launches;
    info.matvecs += cr.matvecs;
    int dmax = 0, dmin = 1 << 30;
    for (int d : cr.depth) { dmax = std::max(dmax, d); dmin = std::min(dmin, d); }
    info.cf_depth_max = dmax;
    info.cf_depth_min = dmin;
    info.seconds_second_step = secs(t0);
    info.seconds_total = secs(t_start);
    info.kernel_launches = launches;
    if (sr.status == MSB_EMAXITER) fail(MSB_EMAXITER, "some incident energies did not converge (maps written)");
}

}  // namespace msb

static bool same_model(const msb_model& a, const msb_model& b) {
    return a.L == b.L && a.n_up == b.n_up && a.n_dn == b.n_dn && a.periodic == b.periodic && a.t == b.t &&
           a.U == b.U && a.Uc == b.Uc && a.core_site == b.core_site && a.o2_spin == b.o2_spin &&
           a.o1_spin == b.o1_spin && a.lx == b.lx && a.tp == b.tp;
}

extern "C" msb_status msb_rixs_map_ops(msb_op* H, msb_op* Hp, const msb_map_params* params, const double* G,
                                       double E_G, const double* w_in, int n_in, const double* w, int n_w,
                                       double* I_dev, msb_solve_info* info, void* stream) {
    if (info) *info = msb_solve_info{};
    return msb::guard("msb_rixs_map_ops", [&] {
        msb::require_device();
        MSB_REQUIRE(H != nullptr && Hp != nullptr && params != nullptr, "NULL argument");
        MSB_REQUIRE(H->kind == 0 && Hp->kind == 0 && H->intermediate == 0 && Hp->intermediate == 1,
                    "H and Hp must be the Hubbard operators of one model (sectors 0 and 1)");
        MSB_REQUIRE(same_model(H->model, Hp->model), "H and Hp belong to different models");
        msb::g_alloc_bytes = 0;
        msb_solve_info local{};
        msb::StreamScope scope((cudaStream_t)stream);
        struct Fill {
            msb_solve_info* dst; msb_solve_info* src;
            ~Fill() { if (dst) { src->device_bytes = msb::g_alloc_bytes; *dst = *src; } }
        } fill{info, &local};
        msb::rixs_map_core(H, Hp, H->model, *params, G, E_G, w_in, n_in, w, n_w, I_dev, true, local, scope.s, 0);
        scope.finish();
        msb::prof_collect();
    });
}

extern "C" msb_status msb_rixs_map_sites(const msb_model* model, const msb_map_params* params, const int* sites,
                                         int n_sites, const double* w_in, int n_in, const double* w, int n_w,
                                         double* I_out, msb_solve_info* info, void* stream) {
    if (info) *info = msb_solve_info{};
    return msb::guard("msb_rixs_map_sites", [&] {
        msb::require_device();
        MSB_REQUIRE(model != nullptr && params != nullptr, "NULL argument");
        msb::g_alloc_bytes = 0;
        msb_solve_info local{};
        msb::StreamScope scope((cudaStream_t)stream);
        struct Fill {
            msb_solve_info* dst; msb_solve_info* src;
            ~Fill() { if (dst) { src->device_bytes = msb::g_alloc_bytes; *dst = *src; } }
        } fill{info, &local};
        msb::rixs_map_sites_impl(*model, *params, sites, n_sites, w_in, n_in, w, n_w, I_out, local, scope.s);
        scope.finish();
        msb::prof_collect();
    });
}

extern "C" msb_status msb_rixs_map_q(const msb_model* model, const msb_map_params* params, const double* qs, int n_q,
                                     const double* w_in, int n_in, const double* w, int n_w, double* I_out,
                                     msb_solve_info* info, void* stream) {
    if (info) *info = msb_solve_info{};
    return msb::guard("msb_rixs_map_q", [&] {
        msb::require_device();
        MSB_REQUIRE(model != nullptr && params != nullptr && qs != nullptr, "NULL argument");
        MSB_REQUIRE(n_q >= 1 && int64_t(n_q) * n_in <= 65535, "need 1 <= n_q and n_q * n_in <= 65535");
        for (int q = 0; q < n_q; ++q) MSB_REQUIRE(std::isfinite(qs[q]), "momenta must be finite");
        msb::validate_model(*model);
        std::vector<int> sites(model->L);
        for (int j = 0; j < model->L; ++j) sites[j] = j;
        msb::g_alloc_bytes = 0;
        msb_solve_info local{};
        msb::StreamScope scope((cudaStream_t)stream);
        struct Fill {
            msb_solve_info* dst; msb_solve_info* src;
            ~Fill() { if (dst) { src->device_bytes = msb::g_alloc_bytes; *dst = *src; } }
        } fill{info, &local};
        msb::rixs_map_sites_impl(*model, *params, sites.data(), model->L, w_in, n_in, w, n_w, I_out, local, scope.s,
                                 qs, n_q);
        scope.finish();
        msb::prof_collect();
    });
}

extern "C" msb_status msb_rixs_map(const msb_model* model, const msb_map_params* params, const double* G, double E_G,
                                   const double* w_in, int n_in, const double* w, int n_w, double* I_out,
                                   msb_solve_info* info, void* stream) {
    if (info) *info = msb_solve_info{};
    return msb::guard("msb_rixs_map", [&] {
        msb::require_device();
        MSB_REQUIRE(model != nullptr && params != nullptr, "NULL argument");
        msb::g_alloc_bytes = 0;
        msb_solve_info local{};
        msb::StreamScope scope((cudaStream_t)stream);
        struct Fill {
            msb_solve_info* dst; msb_solve_info* src;
            ~Fill() { if (dst) { src->device_bytes = msb::g_alloc_bytes; *dst = *src; } }
        } fill{info, &local};
        msb::rixs_map(*model, *params, G, E_G, w_in, n_in, w, n_w, I_out, local, scope.s);
        scope.finish();
        msb::prof_collect();
    });
}

extern "C" msb_status msb_rixs_map_clusters(const msb_model* models, int n_clusters, const msb_map_params* params,
                                            const double* w_in, int n_in, const double* w, int n_w, double* I_out,
                                            double* E_G_out, msb_solve_info* info, void* stream) {
    if (info) *info = msb_solve_info{};
    return msb::guard("msb_rixs_map_clusters", [&] {
        msb::require_device();
        MSB_REQUIRE(models != nullptr && params != nullptr, "NULL argument");
        msb::g_alloc_bytes = 0;
        msb_solve_info local{};
        msb::StreamScope scope((cudaStream_t)stream);
        struct Fill {
            msb_solve_info* dst; msb_solve_info* src;
            ~Fill() { if (dst) { src->device_bytes = msb::g_alloc_bytes; *dst = *src; } }
        } fill{info, &local};
        msb::rixs_map_clusters_impl(models, n_clusters, *params, w_in, n_in, w, n_w, I_out, E_G_out, local, scope.s);
        scope.finish();
        msb::prof_collect();
    });
}
