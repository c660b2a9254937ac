// Operator objects and the plain apply y = (A + c0) x (the MVM of Alg. 1).
#include <cmath>
#include <memory>

#include "operator.cuh"
#include "kernels.cuh"
#include "profile.cuh"

namespace msb {

// Electron counts of the model's sectors: 0 ground, 1 intermediate (after O2 =
// c^dag_{j,o2_spin}), 2 final (after O1 = c_{j,o1_spin}).
void model_sector(const msb_model& m, int which, int& n_up, int& n_dn) {
    n_up = m.n_up;
    n_dn = m.n_dn;
    if (which >= 1) (m.o2_spin == 0 ? n_up : n_dn) += 1;
    if (which == 2) (m.o1_spin == 0 ? n_up : n_dn) -= 1;
}

static void build_hubbard(msb_op* op, const msb_model& m, int intermediate) {
    validate_model(m);
    MSB_REQUIRE(intermediate >= 0 && intermediate <= 2, "sector must be 0 (ground), 1 (intermediate) or 2 (final)");
    int nu = 0, nd = 0;
    model_sector(m, intermediate, nu, nd);
    MSB_REQUIRE(nu >= 0 && nu <= m.L && nd >= 0 && nd <= m.L, "the sector's electron counts must be in 0..L");
    op->kind = 0;
    op->model = m;
    op->intermediate = intermediate;
    op->sec_up = nu;
    op->sec_dn = nd;
    op->host_up = sector_states(m.L, op->sec_up);
    op->host_dn = sector_states(m.L, op->sec_dn);
    std::vector<int32_t> tu, td;
    std::vector<uint8_t> cu, cd;
    int Wu = 0, Wd = 0;
    std::vector<uint8_t> du, dd;
    const bool flux = m.flux != 0.0;
    hop_table(m.L, op->sec_up, m.periodic != 0, op->host_up, tu, cu, Wu, m.lx, flux ? &du : nullptr);
    hop_table(m.L, op->sec_dn, m.periodic != 0, op->host_dn, td, cd, Wd, m.lx, flux ? &dd : nullptr);
    if (flux) {
        op->dirup.alloc(du.size()); op->dirup.upload(du.data(), du.size());
        op->dirdn.alloc(dd.size()); op->dirdn.upload(dd.data(), dd.size());
    }
    if (m.lx > 0 && m.tp != 0.0) {
        const auto bonds = lattice_bonds(m.L, true, m.lx, true);
        std::vector<int32_t> tu2, td2;
        std::vector<uint8_t> cu2, cd2;
        int Wu2 = 0, Wd2 = 0;
        hop_table_bonds(bonds, 1, m.L, op->sec_up, op->host_up, tu2, cu2, Wu2);
        hop_table_bonds(bonds, 1, m.L, op->sec_dn, op->host_dn, td2, cd2, Wd2);
        op->hup2.alloc(tu2.size()); op->hup2.upload(tu2.data(), tu2.size());
        op->hdn2.alloc(td2.size()); op->hdn2.upload(td2.data(), td2.size());
        op->nup2.alloc(cu2.size()); op->nup2.upload(cu2.data(), cu2.size());
        op->ndn2.alloc(cd2.size()); op->ndn2.upload(cd2.data(), cd2.size());
        op->hub.Wup2 = Wu2;
        op->hub.Wdn2 = Wd2;
        double nh2 = 0;
        for (uint8_t c : cu2) nh2 += double(c) * double(cd.size());
        for (uint8_t c : cd2) nh2 += double(c) * double(cu.size());
        op->offdiag2 = nh2;
    }
    MSB_CUDA(cudaGetDevice(&op->device));
    op->hup.alloc(tu.size()); op->hup.upload(tu.data(), tu.size());
    op->hdn.alloc(td.size()); op->hdn.upload(td.data(), td.size());
    op->nup.alloc(cu.size()); op->nup.upload(cu.data(), cu.size());
    op->ndn.alloc(cd.size()); op->ndn.upload(cd.data(), cd.size());
    op->sup.alloc(op->host_up.size()); op->sup.upload(op->host_up.data(), op->host_up.size());
    op->sdn.alloc(op->host_dn.size()); op->sdn.upload(op->host_dn.data(), op->host_dn.size());
    if (op->host_dn.size() < 32768) {
        // position-indexed copies for the continued fraction's row order
        const int64_t D = int64_t(op->host_dn.size());
        const std::vector<uint16_t>& ord = cached_row_order(m.L, op->sec_dn, m.periodic != 0, m.lx);
        MSB_REQUIRE(int64_t(ord.size()) == D, "row order size mismatch");
        std::vector<int32_t> tpos;
        std::vector<uint8_t> cpos;
        table_in_row_order(td, cd, D, Wd, ord, tpos, cpos);
        std::vector<uint32_t> spos(static_cast<size_t>(D));
        for (int64_t p = 0; p < D; ++p) spos[p] = op->host_dn[ord[p]];
        op->dpos.alloc(ord.size()); op->dpos.upload(ord.data(), ord.size());
        op->ndnp.alloc(cpos.size()); op->ndnp.upload(cpos.data(), cpos.size());
        op->sdnp.alloc(spos.size()); op->sdnp.upload(spos.data(), spos.size());
        std::vector<uint16_t> t16(tpos.size());
        // empty slots point at index Ddn, where the row-tiled apply keeps a zero
        const uint16_t empty = uint16_t(D << 1);
        for (size_t i = 0; i < tpos.size(); ++i) t16[i] = tpos[i] < 0 ? empty : uint16_t(tpos[i]);
        op->hdn16.alloc(t16.size());
        op->hdn16.upload(t16.data(), t16.size());
        if (D % 2 == 0 && D >= 2 && D + kRowZeroWords < 32768) {
            // targets moved to their shared-memory slots, hops in their scheduled rounds,
            // for the FP32 row-tiled apply
            const RowLayout& lay = cached_row_layout(m.L, op->sec_dn, m.periodic != 0, kApplyThreads, m.lx);
            MSB_REQUIRE(int64_t(lay.perm.size()) == D, "row layout size mismatch");
            // entries in the layout's round order (the same hops per position)
            MSB_REQUIRE(lay.table.size() == tpos.size(), "row schedule size mismatch");
            std::vector<uint16_t> tp(tpos.size());
            for (size_t i = 0; i < tpos.size(); ++i) {
                const int32_t e = lay.table[i];
                const int32_t t = e >> 1;
                MSB_REQUIRE(t >= 0 && t < D + kRowZeroWords, "hop target out of range");
                tp[i] = t >= D ? uint16_t(e) : uint16_t((int32_t(lay.perm[t]) << 1) | (e & 1));   // zero words stay
            }
            op->hdn16p.alloc(tp.size());
            op->hdn16p.upload(tp.data(), tp.size());
            op->slot16.alloc(lay.perm.size());
            op->slot16.upload(lay.perm.data(), lay.perm.size());
        }
    }
    MSB_CUDA(cudaDeviceSynchronize());
    HubView& h = op->hub;
    h.Dup = int64_t(op->host_up.size());
    h.Ddn = int64_t(op->host_dn.size());
    h.Wup = Wu;
    h.Wdn = Wd;
    h.hup = op->hup.p; h.hdn = op->hdn.p;
    h.nup = op->nup.p; h.ndn = op->ndn.p;
    h.dpos = op->dpos.p;
    h.ndnp = op->ndnp.p;
    h.sdnp = op->sdnp.p;
    h.hdn16 = op->hdn16.p;
    h.hdn16p = op->hdn16p.p;
    h.slot16 = op->slot16.p;
    h.sup = op->sup.p; h.sdn = op->sdn.p;
    {
        bool un = false, dn = false;
        for (int32_t e : tu) un = un || (e >= 0 && (e & 1));
        for (int32_t e : td) dn = dn || (e >= 0 && (e & 1));
        h.usign = un ? 1 : 0;
        h.dsign = dn ? 1 : 0;
    }
    h.t = m.t; h.U = m.U; h.Uc = m.Uc;
    h.hup2 = op->hup2.p; h.hdn2 = op->hdn2.p;
    h.nup2 = op->nup2.p; h.ndn2 = op->ndn2.p;
    h.t2 = m.tp;
    h.dirup = op->dirup.p;
    h.dirdn = op->dirdn.p;
    h.cth = std::cos(m.flux / m.L);
    h.sth = std::sin(m.flux / m.L);
    h.tf = float(m.t); h.Uf = float(m.U); h.Ucf = float(m.Uc);
    h.core = intermediate == 1 ? m.core_site : -1;
    h.L = m.L;
    op->dim = h.Dup * h.Ddn;
    double nh = 0;
    for (uint8_t c : cu) nh += double(c) * double(h.Ddn);
    for (uint8_t c : cd) nh += double(c) * double(h.Dup);
    op->offdiag = nh + op->offdiag2;
}

static void build_csr(msb_op* op, int64_t n, const int64_t* rowptr, const int32_t* col,
                      const double* val) {
    MSB_REQUIRE(n > 0 && rowptr && col && val, "invalid CSR arguments");
    MSB_REQUIRE(rowptr[0] == 0, "rowptr[0] must be 0");
    const int64_t nnz = rowptr[n];
    MSB_REQUIRE(nnz >= 0, "rowptr[n] must be >= 0");
    for (int64_t i = 0; i < n; ++i) MSB_REQUIRE(rowptr[i + 1] >= rowptr[i], "rowptr must be non-decreasing");
    for (int64_t k = 0; k < nnz; ++k) MSB_REQUIRE(col[k] >= 0 && col[k] < n, "column index out of range");
    op->kind = 1;
    op->dim = n;
    MSB_CUDA(cudaGetDevice(&op->device));
    op->rowptr.alloc(size_t(n + 1)); op->rowptr.upload(rowptr, size_t(n + 1));
    op->col.alloc(size_t(nnz)); op->col.upload(col, size_t(nnz));
    op->val64.alloc(size_t(nnz)); op->val64.upload(val, size_t(nnz));
    std::vector<float> v32(val, val + nnz);
    for (int64_t k = 0; k < nnz; ++k) v32[k] = float(val[k]);
    op->val32.alloc(size_t(nnz)); op->val32.upload(v32.data(), size_t(nnz));
    MSB_CUDA(cudaDeviceSynchronize());
    op->csr = CsrView{n, op->rowptr.p, op->col.p, op->val64.p, op->val32.p};
    op->offdiag = double(nnz);
}

static void build_sum(msb_op* op, const msb_op* const* ops, const double* shifts, int n) {
    MSB_REQUIRE(ops != nullptr && n >= 1 && n <= kMaxParts, "need 1..16 operators");
    op->kind = 2;
    SumView& v = op->sum;
    v.np = n;
    int64_t off = 0;
    MSB_CUDA(cudaGetDevice(&op->device));
    for (int i = 0; i < n; ++i) {
        MSB_REQUIRE(ops[i] != nullptr && ops[i]->kind == 0, "every part must be a Hubbard operator");
        MSB_REQUIRE(ops[i]->device == op->device, "every part must live on the current device");
        v.part[i] = ops[i]->hub;
        v.off[i] = off;
        v.shift[i] = shifts ? shifts[i] : 0.0;
        MSB_REQUIRE(std::isfinite(v.shift[i]), "shifts must be finite");
        off += ops[i]->dim;
        op->offdiag += ops[i]->offdiag;
        op->parts.push_back(ops[i]);
    }
    for (int i = n; i <= kMaxParts; ++i) v.off[i] = off;
    op->dim = off;
}

// ---------------------------------------------------------------------------
// y_c = (A + c0) x_c for every column c = blockIdx.y.
// ---------------------------------------------------------------------------
template <class View, typename V>
__global__ void __launch_bounds__(256) k_apply(View op, const V* __restrict__ x, V* __restrict__ y,
                                               int64_t n, double c0r, double c0i) {
    const V* __restrict__ xc = x + int64_t(blockIdx.y) * n;
    V* __restrict__ yc = y + int64_t(blockIdx.y) * n;
    for (int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; s < n;
         s += int64_t(gridDim.x) * blockDim.x) {
        const V xs = xc[s];
        const V h = op.hx(s, xc, xs);
        yc[s] = vadd(h, cscale(c0r, c0i, xs));
    }
}

template <class View>
static void launch_apply(const msb_op* op, const View& v, int64_t n, double2 c0, const void* x, void* y, int nvec,
                         msb_precision prec, cudaStream_t st) {
    dim3 grid(grid_for(n, 256, 8), nvec);
    const size_t csz = prec == MSB_FP64 ? 16 : 8;
    ProfScope ps("h_apply", st, nvec * (2.0 * n * csz + op->matrix_bytes(csz)), nvec * (op->hx_flops() + 8.0 * n));
    if (prec == MSB_FP64)
        k_apply<View, double2><<<grid, 256, 0, st>>>(v, (const double2*)x, (double2*)y, n, c0.x, c0.y);
    else
        k_apply<View, float2><<<grid, 256, 0, st>>>(v, (const float2*)x, (float2*)y, n, c0.x, c0.y);
    MSB_LAUNCH_CHECK();
    count_launch();
}

void op_apply(msb_op* op, double2 c0, const void* x, void* y, int nvec, msb_precision prec,
              cudaStream_t st) {
    MSB_REQUIRE(op != nullptr, "operator is NULL");
    MSB_REQUIRE(x != nullptr && y != nullptr, "x / y is NULL");
    MSB_REQUIRE(nvec >= 1 && nvec <= 65535, "nvec must be in 1..65535");
    MSB_REQUIRE(prec == MSB_FP64 || prec == MSB_FP32_MIXED, "unknown precision");
    if (op->kind == 0) launch_apply(op, op->hub, op->dim, c0, x, y, nvec, prec, st);
    else if (op->kind == 1) launch_apply(op, op->csr, op->dim, c0, x, y, nvec, prec, st);
    else launch_apply(op, op->sum, op->dim, c0, x, y, nvec, prec, st);
    prof_collect();
}

}  // namespace msb

// ----------------------------------------------------------------------------
// C ABI: operators
// ----------------------------------------------------------------------------
extern "C" msb_status msb_op_create_hubbard(const msb_model* model, int intermediate, msb_op** out) {
    return msb::guard("msb_op_create_hubbard", [&] {
        MSB_REQUIRE(model != nullptr && out != nullptr, "NULL argument");
        msb::require_device();
        auto op = std::make_unique<msb_op>();
        msb::build_hubbard(op.get(), *model, intermediate);
        *out = op.release();
    });
}

extern "C" msb_status msb_op_create_csr(int64_t n, const int64_t* rowptr, const int32_t* col,
                                        const double* val, msb_op** out) {
    return msb::guard("msb_op_create_csr", [&] {
        MSB_REQUIRE(out != nullptr, "out is NULL");
        msb::require_device();
        auto op = std::make_unique<msb_op>();
        msb::build_csr(op.get(), n, rowptr, col, val);
        *out = op.release();
    });
}

extern "C" msb_status msb_op_create_direct_sum(const msb_op* const* ops, const double* shifts, int n,
                                               msb_op** out) {
    return msb::guard("msb_op_create_direct_sum", [&] {
        MSB_REQUIRE(out != nullptr, "out is NULL");
        msb::require_device();
        auto op = std::make_unique<msb_op>();
        msb::build_sum(op.get(), ops, shifts, n);
        *out = op.release();
    });
}

extern "C" msb_status msb_op_dim(const msb_op* op, int64_t* dim) {
    return msb::guard("msb_op_dim", [&] {
        MSB_REQUIRE(op != nullptr && dim != nullptr, "NULL argument");
        *dim = op->dim;
    });
}

extern "C" void msb_op_destroy(msb_op* op) { delete op; }

extern "C" msb_status msb_op_apply(msb_op* op, msb_complex c0, const void* x, void* y, int nvec,
                                   msb_precision prec, void* stream) {
    return msb::guard("msb_op_apply", [&] {
        msb::require_device();
        msb::op_apply(op, make_double2(c0.re, c0.im), x, y, nvec, prec, (cudaStream_t)stream);
    });
}
