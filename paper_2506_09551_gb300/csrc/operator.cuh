// Operators of the solver: the matrix-free Hubbard Hamiltonian H / H'
// (Eqs. 9-10) on a bit-string sector basis, and a general real symmetric CSR
// matrix.  Both expose a device "view" with one method,
//     V hx(s, x, xs)  =  (A x)[s]      (xs = x[s], already loaded)
// which every apply-style kernel (plain apply, seed MVM with fused bilinear
// product, Lanczos step with fused Hermitian product) calls per element.
#pragma once

#include <type_traits>

#include "common.cuh"

namespace msb {

// ---- value-type helpers: V is double, float (real vectors) or double2,
// float2 (complex vectors); S is the matching real scalar. ----
__device__ __forceinline__ double vzero(double) { return 0.0; }
__device__ __forceinline__ float vzero(float) { return 0.0f; }
__device__ __forceinline__ double2 vzero(double2) { return make_double2(0.0, 0.0); }
__device__ __forceinline__ float2 vzero(float2) { return make_float2(0.f, 0.f); }
__device__ __forceinline__ double vadd(double a, double b) { return a + b; }
__device__ __forceinline__ float vadd(float a, float b) { return a + b; }
__device__ __forceinline__ double2 vadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 vadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double vsub(double a, double b) { return a - b; }
__device__ __forceinline__ float vsub(float a, float b) { return a - b; }
__device__ __forceinline__ double2 vsub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 vsub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
// a * v + acc (real a)
__device__ __forceinline__ double vaxpy(double a, double v, double acc) { return fma(a, v, acc); }
__device__ __forceinline__ float vaxpy(float a, float v, float acc) { return fmaf(a, v, acc); }
__device__ __forceinline__ double2 vaxpy(double a, double2 v, double2 acc) {
    return make_double2(fma(a, v.x, acc.x), fma(a, v.y, acc.y));
}
__device__ __forceinline__ float2 vaxpy(float a, float2 v, float2 acc) {
    return make_float2(fmaf(a, v.x, acc.x), fmaf(a, v.y, acc.y));
}
__device__ __forceinline__ double vscale(double a, double v) { return a * v; }
__device__ __forceinline__ float vscale(float a, float v) { return a * v; }
__device__ __forceinline__ double2 vscale(double a, double2 v) { return make_double2(a * v.x, a * v.y); }
__device__ __forceinline__ float2 vscale(float a, float2 v) { return make_float2(a * v.x, a * v.y); }

template <typename V> struct Scalar;
template <> struct Scalar<double> { using type = double; };
template <> struct Scalar<float> { using type = float; };
template <> struct Scalar<double2> { using type = double; };
template <> struct Scalar<float2> { using type = float; };
template <typename V> using scalar_t = typename Scalar<V>::type;
template <typename V>
constexpr bool is_cplx_v = std::is_same<V, double2>::value || std::is_same<V, float2>::value;

// ----------------------------------------------------------------------------
// Hubbard view.  Basis index s = iu * Ddn + id.  Hop tables are ELL with the
// hop slot as the slow index ([slot][state]) so that consecutive threads
// (consecutive id) read consecutive entries.  An entry is
// (target_rank << 1) | (sign < 0), -1 when empty; valid entries come first
// and n{up,dn}[state] counts them.  The matrix element of a hop is -t * sign.
// ----------------------------------------------------------------------------
struct HubView {
    int64_t Dup, Ddn;
    int Wup, Wdn;
    const int32_t* hup;
    const int32_t* hdn;
    const uint8_t* nup;
    const uint8_t* ndn;
    // Continued-fraction row order (Ddn < 32768, else all null): the row-tiled
    // apply kernels hold position p of a row as down state dpos[p] (states
    // sorted by hop count) and use these position-indexed arrays.
    const uint16_t* dpos;   // down state at position p
    const uint8_t* ndnp;    // its hop count
    const uint32_t* sdnp;   // its occupation string
    const uint16_t* hdn16;  // [slot][position] down-spin table, entries (target position << 1) | neg;
                            // empty slots hold Ddn << 1 (index Ddn: a zero kept past the staged row)
    const uint16_t* hdn16p; // the same with targets moved to their shared-memory slots (FP32 apply), or null
    const uint16_t* slot16; // shared-memory slot of each position (with hdn16p), or null
    const uint32_t* sup;   // occupation strings, rank order
    const uint32_t* sdn;
    int usign, dsign;      // 1 if some up / down hop carries a negative sign (Jordan-Wigner string)
    // diagonal bonds of a 2D cluster (hopping t2 = t'), same layout; null without them
    int Wup2, Wdn2;
    const int32_t* hup2;
    const int32_t* hdn2;
    const uint8_t* nup2;
    const uint8_t* ndn2;
    double t2;
    // Peierls phases (flux through the ring): per hop entry 1 if the hop carries
    // exp(+i theta), 0 for exp(-i theta); null without a flux
    const uint8_t* dirup;
    const uint8_t* dirdn;
    double cth, sth;       // cos theta, sin theta, theta = flux / L
    double t, U, Uc;
    int core;              // core-hole site, -1: none (plain H)
    int L;                 // sites
    float tf, Uf, Ucf;     // t, U, Uc rounded to FP32 (FP32 kernels use no FP64 arithmetic)

    // U popc(u & d) - Uc (n_{j,up} + n_{j,dn}), in the vector's precision (no
    // FP64 work in the FP32 path).
    template <typename S>
    __device__ __forceinline__ S diag(int64_t iu, int64_t id) const {
        const uint32_t a = __ldg(sup + iu), b = __ldg(sdn + id);
        S v = S(U) * S(__popc(a & b));
        if (core >= 0) v -= S(Uc) * S(((a >> core) & 1u) + ((b >> core) & 1u));
        return v;
    }

    // Hopping sum with the Peierls phase of every hop (complex vectors only).
    template <typename V>
    __device__ __forceinline__ V hop_sum_phased(int64_t iu, int64_t id, const V* __restrict__ x) const {
        using S = scalar_t<V>;
        S ar = 0, ai = 0;
        const S c = S(cth), s = S(sth);
        const int nu = __ldg(nup + iu);
        for (int e = 0; e < nu; ++e) {
            const int32_t h = __ldg(hup + int64_t(e) * Dup + iu);
            const V v = x[int64_t(h >> 1) * Ddn + id];
            const S sg = (h & 1) ? S(-1) : S(1), ss = __ldg(dirup + int64_t(e) * Dup + iu) ? s : -s;
            ar += sg * (c * v.x - ss * v.y);
            ai += sg * (c * v.y + ss * v.x);
        }
        const int nd = __ldg(ndn + id);
        const V* __restrict__ xrow = x + iu * Ddn;
        for (int e = 0; e < nd; ++e) {
            const int32_t h = __ldg(hdn + int64_t(e) * Ddn + id);
            const V v = xrow[h >> 1];
            const S sg = (h & 1) ? S(-1) : S(1), ss = __ldg(dirdn + int64_t(e) * Ddn + id) ? s : -s;
            ar += sg * (c * v.x - ss * v.y);
            ai += sg * (c * v.y + ss * v.x);
        }
        return mk(ar, ai);
    }

    template <typename V>
    __device__ __forceinline__ V hx_at(int64_t iu, int64_t id, const V* __restrict__ x, V xs) const {
        using S = scalar_t<V>;
        if constexpr (is_cplx_v<V>) {
            if (dirup) return vaxpy(S(-t), hop_sum_phased(iu, id, x), vscale(diag<S>(iu, id), xs));
        }
        V acc = vzero(xs);
        const int nu = __ldg(nup + iu);
        for (int e = 0; e < nu; ++e) {
            const int32_t h = __ldg(hup + int64_t(e) * Dup + iu);
            const V v = x[int64_t(h >> 1) * Ddn + id];
            acc = (h & 1) ? vsub(acc, v) : vadd(acc, v);
        }
        const int nd = __ldg(ndn + id);
        const V* __restrict__ xrow = x + iu * Ddn;
        for (int e = 0; e < nd; ++e) {
            const int32_t h = __ldg(hdn + int64_t(e) * Ddn + id);
            const V v = xrow[h >> 1];
            acc = (h & 1) ? vsub(acc, v) : vadd(acc, v);
        }
        // H x = diag * x - t * sum(sign * x_neighbour) - t2 * sum over the diagonal bonds
        V out = vaxpy(S(-t), acc, vscale(diag<S>(iu, id), xs));
        if (hup2) {
            V acc2 = vzero(xs);
            const int nu2 = __ldg(nup2 + iu);
            for (int e = 0; e < nu2; ++e) {
                const int32_t h = __ldg(hup2 + int64_t(e) * Dup + iu);
                const V v = x[int64_t(h >> 1) * Ddn + id];
                acc2 = (h & 1) ? vsub(acc2, v) : vadd(acc2, v);
            }
            const int nd2 = __ldg(ndn2 + id);
            for (int e = 0; e < nd2; ++e) {
                const int32_t h = __ldg(hdn2 + int64_t(e) * Ddn + id);
                const V v = xrow[h >> 1];
                acc2 = (h & 1) ? vsub(acc2, v) : vadd(acc2, v);
            }
            out = vaxpy(S(-t2), acc2, out);
        }
        return out;
    }

    template <typename V>
    __device__ __forceinline__ V hx(int64_t s, const V* __restrict__ x, V xs) const {
        const int64_t iu = s / Ddn, id = s - iu * Ddn;
        return hx_at(iu, id, x, xs);
    }
};

// ----------------------------------------------------------------------------
// Direct sum of Hubbard operators (block diagonal): element s in
// [off[i], off[i+1]) belongs to part i, and (A x)[s] = (H_i x_i)[s - off[i]]
// + shift[i] x[s].  One launch over the concatenated vector applies every part,
// so one Krylov recurrence serves independent clusters of uneven size.
// ----------------------------------------------------------------------------
constexpr int kMaxParts = 16;

struct SumView {
    int np;
    int64_t off[kMaxParts + 1];
    double shift[kMaxParts];
    HubView part[kMaxParts];

    template <int I, typename V>
    __device__ __forceinline__ V hx_part(int64_t s, const V* __restrict__ x, V xs) const {
        using S = scalar_t<V>;
        const V h = part[I].hx(s - off[I], x + off[I], xs);
        return vaxpy(S(shift[I]), xs, h);
    }

    template <typename V>
    __device__ __forceinline__ V hx(int64_t s, const V* __restrict__ x, V xs) const {
        // part index by comparison with constant indices (no dynamic indexing of the
        // parameter arrays), then a switch on it
        int i = 0;
#pragma unroll
        for (int j = 1; j < kMaxParts; ++j)
            if (j < np && s >= off[j]) i = j;
        switch (i) {
#define MSB_SUM_CASE(I) case I: return hx_part<I>(s, x, xs);
            MSB_SUM_CASE(1) MSB_SUM_CASE(2) MSB_SUM_CASE(3) MSB_SUM_CASE(4) MSB_SUM_CASE(5) MSB_SUM_CASE(6)
            MSB_SUM_CASE(7) MSB_SUM_CASE(8) MSB_SUM_CASE(9) MSB_SUM_CASE(10) MSB_SUM_CASE(11) MSB_SUM_CASE(12)
            MSB_SUM_CASE(13) MSB_SUM_CASE(14) MSB_SUM_CASE(15)
#undef MSB_SUM_CASE
            default: return hx_part<0>(s, x, xs);
        }
    }
};

// ----------------------------------------------------------------------------
// CSR view of a real symmetric matrix (val in the vector's scalar precision).
// ----------------------------------------------------------------------------
struct CsrView {
    int64_t n;
    const int64_t* rowptr;
    const int32_t* col;
    const double* val64;
    const float* val32;

    template <typename V>
    __device__ __forceinline__ V hx(int64_t s, const V* __restrict__ x, V xs) const {
        using S = scalar_t<V>;
        V acc = vzero(xs);
        const int64_t b = __ldg(rowptr + s), e = __ldg(rowptr + s + 1);
        if constexpr (sizeof(S) == 8) {
            for (int64_t k = b; k < e; ++k) acc = vaxpy(__ldg(val64 + k), x[__ldg(col + k)], acc);
        } else {
            for (int64_t k = b; k < e; ++k) acc = vaxpy(__ldg(val32 + k), x[__ldg(col + k)], acc);
        }
        return acc;
    }
};

}  // namespace msb

// ----------------------------------------------------------------------------
// Library-side operator object (host).
// ----------------------------------------------------------------------------
struct msb_op {
    int kind = 0;                // 0 Hubbard, 1 CSR, 2 direct sum of Hubbard operators
    int64_t dim = 0;
    // Hubbard
    msb_model model{};
    int intermediate = 0;
    int sec_up = 0, sec_dn = 0;  // electrons of this operator's sector
    msb::DevBuf<int32_t> hup, hdn, hup2, hdn2;
    msb::DevBuf<uint8_t> dirup, dirdn;
    msb::DevBuf<uint8_t> nup, ndn, nup2, ndn2;
    msb::DevBuf<uint16_t> hdn16, hdn16p, slot16, dpos;
    msb::DevBuf<uint8_t> ndnp;
    msb::DevBuf<uint32_t> sdnp;
    msb::DevBuf<uint32_t> sup, sdn;
    std::vector<uint32_t> host_up, host_dn;
    msb::HubView hub{};
    // CSR
    msb::DevBuf<int64_t> rowptr;
    msb::DevBuf<int32_t> col;
    msb::DevBuf<double> val64;
    msb::DevBuf<float> val32;
    msb::CsrView csr{};
    // direct sum (parts are not owned: the caller keeps them alive)
    std::vector<const msb_op*> parts;
    msb::SumView sum{};
    int device = 0;
    double offdiag = 0;          // off-diagonal entries (hops, or CSR nonzeros)
    double offdiag2 = 0;         // of them, the diagonal-bond hops of a 2D cluster

    // Floating-point operations of one application (A x)[all s] on complex
    // vectors: two adds per hop plus the diagonal and hopping scale (Hubbard),
    // or a complex-by-real multiply-add per nonzero (CSR).  Halve for real vectors.
    double hx_flops() const { return kind != 1 ? 2.0 * offdiag + 6.0 * double(dim) : 4.0 * offdiag; }
    // Bytes of the matrix itself read by one application (zero when matrix-free).
    double matrix_bytes(size_t csz) const {
        return kind != 1 ? 0.0 : offdiag * (4.0 + (csz == 16 ? 8.0 : 4.0)) + double(dim + 1) * 8.0;
    }
};

namespace msb {
// Threads per CTA of the row-tiled continued-fraction apply kernels.
constexpr int kApplyThreads = 256;
// Zero words kept past a row staged in shared memory by the FP32 row-tiled
// apply, one on each of the 16 bank pairs (idle hop rounds read one of them).
constexpr int kRowZeroWords = 16;
// Shared-memory slot of each down-spin position and the round of each of its
// hops for the FP32 row-tiled apply (basis.cu): perm[p] = slot of position p;
// table[k * D + p] = the position-space entry (target << 1 | sign) position p
// reads in round k, a target D + b naming zero word b; costs = mean worst-bank count per
// half-warp gather, identity slots in hop order and the chosen layout.
struct RowLayout {
    std::vector<uint16_t> perm;
    std::vector<int32_t> table;
    int width = 0;
    double cost_plain = 0, cost_layout = 0;
};
RowLayout row_layout(const std::vector<int32_t>& table, const std::vector<uint8_t>& count, int64_t D, int W,
                     int threads);
const RowLayout& cached_row_layout(int L, int n, bool periodic, int threads, int lx = 0);
// Continued-fraction row order (basis.cu): order[p] = down state at position p
// of a row, sorted by hop count; the rank-space table rewritten to positions.
std::vector<uint16_t> row_order(const std::vector<uint8_t>& count);
const std::vector<uint16_t>& cached_row_order(int L, int n, bool periodic, int lx = 0);
void table_in_row_order(const std::vector<int32_t>& table, const std::vector<uint8_t>& count, int64_t D, int W,
                        const std::vector<uint16_t>& ord, std::vector<int32_t>& tpos, std::vector<uint8_t>& cpos);
// Host-side sector enumeration and hopping tables (basis.cu).
std::vector<uint32_t> sector_states(int L, int n);
// A bond (i, j) of the lattice; cls 0: hopping t, cls 1: the diagonal hopping t'.
struct Bond { int i, j, cls; };
// Bonds of the chain (lx = 0) or of the periodic lx x (L / lx) cluster (diagonal
// bonds only with diag).
std::vector<Bond> lattice_bonds(int L, bool periodic, int lx, bool diag);
// ELL hop table [W][D] of the class-cls bonds, entries (target << 1) | neg, -1
// empty; counts per state.
// dir (optional): per entry 1 if <state|H|target> moves the electron along the
// bond's direction (i -> j), for the Peierls phase of a flux.
void hop_table_bonds(const std::vector<Bond>& bonds, int cls, int L, int n, const std::vector<uint32_t>& states,
                     std::vector<int32_t>& table, std::vector<uint8_t>& count, int& W,
                     std::vector<uint8_t>* dir = nullptr);
// The nearest-neighbour table of the chain or 2D cluster.
void hop_table(int L, int n, bool periodic, const std::vector<uint32_t>& states,
               std::vector<int32_t>& table, std::vector<uint8_t>& count, int& W, int lx = 0,
               std::vector<uint8_t>* dir = nullptr);
void validate_model(const msb_model& m);
// True for an operator with Peierls phases (complex Hermitian, not complex symmetric).
inline bool op_has_flux(const msb_op* op) {
    if (op->kind == 0) return op->hub.dirup != nullptr;
    if (op->kind == 2) for (const msb_op* q : op->parts) if (q->hub.dirup != nullptr) return true;
    return false;
}
// Electron counts of a model's sector: 0 ground, 1 intermediate, 2 final (operator.cu).
void model_sector(const msb_model& m, int which, int& n_up, int& n_dn);
// y = (A + c0) x for nvec columns (operator.cu).
void op_apply(msb_op* op, double2 c0, const void* x, void* y, int nvec, msb_precision prec,
              cudaStream_t st);
}  // namespace msb
